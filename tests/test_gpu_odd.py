"""GPU tests of the odd-reflection boundary (WAVE2D_BC_ODD): parity against
the FP64 oracle for the Section 6 and derived schemes on every storage type
and one-level kernel, with the difference sums and form, on grids from a few
nodes (several reflections deep) to several tiles; Table 3 reproduced on the
Dirichlet node set; equality with the zero boundary for radius-1 stencils;
bitwise symmetry, checkpoints and the refusals."""
import numpy as np
import pytest

from conftest import load_golden
from gpu_util import TOL, rel_errors, smooth_ic
from initial_data import BC_ODD, BC_ZERO, LAMBDA_MAX, standing_wave_ic
from oracle import derive

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


def _run(w, scheme, u0, v0, h, lam, steps, dtype, kernel, flags=0, bc=BC_ODD):
    ny, nx = u0.shape
    with w.Wave2D(nx, ny, h, lam * h, scheme=scheme, bc=bc, dtype=dtype, flags=flags) as sim:
        sim.set_tuning(kernel=kernel, use_graph=0)
        sim.first_step(u0, v0)
        sim.step_n(steps - 1)
        return sim.get_state()


@pytest.mark.parametrize("scheme", [5, 9, 13])
@pytest.mark.parametrize("dtype,kernel", [(0, 1), (0, 2), (1, 1), (1, 2), (2, 1)],
                         ids=["f64-simple", "f64-tma", "f32-simple", "f32-tma", "f32x2-simple"])
@pytest.mark.parametrize("shape", [(3, 5), (13, 31), (300, 97)], ids=lambda s: f"{s[0]}x{s[1]}")
def test_parity_section6(orc, w, scheme, dtype, kernel, shape):
    nx, ny = shape
    u0, v0, h = smooth_ic(nx, ny, BC_ODD, seed=nx * 3 + scheme)
    lam = 0.9 * LAMBDA_MAX[scheme]
    steps = 40
    up, uc, k = _run(w, scheme, u0, v0, h, lam, steps, dtype, kernel)
    rp, rc, _ = orc.run(scheme, u0, v0, lam, lam * h, steps, bc=BC_ODD)
    assert k == steps
    for got, ref in ((uc, rc), (up, rp)):
        l2, linf = rel_errors(got, ref)
        assert l2 < TOL[dtype] and linf < TOL[dtype], (l2, linf)


@pytest.mark.parametrize("m", [28, 45])
@pytest.mark.parametrize("dtype,kernel,flags", [(0, 2, 0), (1, 1, 0), (1, 2, 0), (1, 2, 4), (1, 2, 8)],
                         ids=["f64-tma", "f32-simple", "f32-tma", "f32-tma-sums", "f32-tma-form"])
@pytest.mark.parametrize("shape", [(5, 7), (150, 77)], ids=lambda s: f"{s[0]}x{s[1]}")
def test_parity_derived(orc, w, m, dtype, kernel, flags, shape):
    nx, ny = shape
    u0, v0, h = smooth_ic(nx, ny, BC_ODD, seed=m + nx)
    s = w.derive_scheme(m)
    lam = 0.9 * w.scheme_lambda_max(s)
    steps = 30
    _, uc, _ = _run(w, s, u0, v0, h, lam, steps, dtype, kernel, flags)
    nodes, wa, wb = derive.node_weights(m, lam)
    _, rc = orc.run_nodes(nodes, wa, wb, u0, v0, lam * h, steps, bc=BC_ODD)
    l2, linf = rel_errors(uc, rc)
    assert l2 < TOL[dtype] and linf < TOL[dtype], (l2, linf)


@pytest.mark.parametrize("flags", [4, 8], ids=["sums", "form"])
def test_parity_difference_variants(orc, w, flags):
    n = 200
    u0, v0, h = smooth_ic(n, 90, BC_ODD, seed=flags)
    lam = 0.9 * LAMBDA_MAX[13]
    _, uc, _ = _run(w, 13, u0, v0, h, lam, 50, w.F32, w.KERNEL_TMA, flags)
    _, rc, _ = orc.run(13, u0, v0, lam, lam * h, 50, bc=BC_ODD)
    l2, linf = rel_errors(uc, rc)
    assert l2 < TOL[1] and linf < TOL[1]


@pytest.mark.parametrize("row", load_golden("table3.txt"), ids=lambda r: f"n{int(r[0])}")
def test_table3_on_the_dirichlet_node_set(w, row):
    """The 13-point standing wave of Table 3 with the odd boundary on the
    nodes 0 < i, j < n, FP64, error tracked by the fused reduction."""
    n, n_t, e_p13, e_c13 = int(row[0]), int(row[1]), row[2], row[3]
    h = 1.0 / n
    u0, v0 = standing_wave_ic(n - 1, n - 1, h, BC_ODD)
    ex = w.exact(w.EXACT_STANDING, amp=1.0, m=1.0, x_off=1.0)
    for flags, printed in ((0, e_p13), (w.CONVENTIONAL, e_c13)):
        with w.Wave2D(n - 1, n - 1, h, 0.707 * h, scheme=13, bc=w.BC_ODD, dtype=w.F64, flags=flags) as sim:
            sim.track_error(ex)
            sim.first_step(u0, v0)
            sim.step_n(n_t - 1)
            _, _, E = sim.error_vs_exact(ex)
        # the printed five digits, up to the GPU's different rounding order
        assert abs(E - printed) <= 1e-4 * printed, (flags, E, printed)


@pytest.mark.parametrize("scheme", [5, 9])
@pytest.mark.parametrize("kernel", [1, 2])
def test_radius_one_equals_zero_boundary_bitwise(w, scheme, kernel):
    n = 130
    u0, v0, h = smooth_ic(n, 70, BC_ZERO, seed=scheme)
    lam = 0.9 * LAMBDA_MAX[scheme]
    a = _run(w, scheme, u0, v0, h, lam, 40, w.F32, kernel, bc=BC_ODD)
    b = _run(w, scheme, u0, v0, h, lam, 40, w.F32, kernel, bc=BC_ZERO)
    assert np.array_equal(a[1], b[1]) and np.array_equal(a[0], b[0])


@pytest.mark.parametrize("kernel", [1, 2])
def test_symmetry_and_kernels_bitwise(w, kernel):
    n = 131
    u0, v0, h = smooth_ic(n, n, BC_ODD, seed=12)
    lam = 0.9 * LAMBDA_MAX[13]
    ref = _run(w, 13, u0, v0, h, lam, 40, w.F32, kernel)[1]
    other = _run(w, 13, u0, v0, h, lam, 40, w.F32, 3 - kernel)[1]
    assert np.array_equal(ref, other)
    for op in (lambda a: np.rot90(a).copy(), lambda a: a.T.copy(), lambda a: a[::-1].copy()):
        assert np.array_equal(_run(w, 13, op(u0), op(v0), h, lam, 40, w.F32, kernel)[1], op(ref))


def test_checkpoint_and_refusals(w):
    n = 64
    u0, v0, h = smooth_ic(n, n, BC_ODD, seed=1)
    with w.Wave2D(n, n, h, 0.5 * h, scheme=13, bc=w.BC_ODD, dtype=w.F32) as a:
        a.first_step(u0, v0)
        a.step_n(20)
        raw, k = a.get_raw()
        a.step_n(30)
        _, ref, _ = a.get_state()
        with pytest.raises(w.Wave2DError) as e:
            a.set_tuning(kernel=w.KERNEL_TEMPORAL)
        assert e.value.code == w.ERR_ARG
        with pytest.raises(w.Wave2DError) as e:
            w.Batch([a])
        assert e.value.code == w.ERR_ARG
    with w.Wave2D(n, n, h, 0.5 * h, scheme=13, bc=w.BC_ODD, dtype=w.F32) as b:
        b.set_raw(raw, k)
        b.step_n(30)
        _, got, _ = b.get_state()
    assert np.array_equal(got, ref)
