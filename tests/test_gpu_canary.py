"""Guard-band canaries (WAVE2D_CANARY) as a stand-in for a memory checker:
every kernel path of the one-level stepping (all schemes, storage types,
boundaries, kernels, difference sums and form), with state loads, raw
checkpoints, norms, error tracking and the autotuner, and the two temporal
kernels on the zero boundary, must leave the NaN pattern in the untouched
part of every plane intact; results stay equal to those of a handle without
canaries."""
import numpy as np
import pytest

from gpu_util import smooth_ic
from initial_data import BC_ODD, BC_PERIODIC, BC_ZERO

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


def _exercise(w, scheme, dtype, bc, kernel, flags, shape):
    nx, ny = shape
    u0, v0, h = smooth_ic(nx, ny, bc, seed=nx + ny)
    lam = 0.5
    out = []
    for extra in (w.CANARY, 0):
        with w.Wave2D(nx, ny, h, lam * h, scheme=scheme, bc=bc, dtype=dtype, flags=flags | extra) as sim:
            sim.set_tuning(kernel=kernel, use_graph=0)
            sim.track_error(w.exact(w.EXACT_NONE))
            sim.first_step(u0, v0)
            sim.step_n(5)                                 # fused tracking kernel
            sim.track_error(None)
            sim.step_n(20)
            sim.error_vs_exact()
            up, uc, k = sim.get_state()
            sim.set_state(up, uc, k)
            sim.step_n(7)
            raw, k = sim.get_raw()
            sim.set_raw(raw, k)
            sim.step_n(7)
            sim.autotune(steps=2)
            sim.set_tuning(kernel=kernel, use_graph=1)
            sim.step_n(40)                                # graph replays
            if extra:
                assert sim.canary_check() == 0
            out.append(sim.get_state()[1])
    assert np.array_equal(out[0], out[1])


CASES = []
for scheme in (5, 9, 13):
    for dtype in (0, 1, 2):
        for bc in (BC_ZERO, BC_PERIODIC, BC_ODD):
            for kernel in ((1,) if dtype == 2 else (1, 2)):
                CASES.append((scheme, dtype, bc, kernel, 0))
    for bc in (BC_ZERO, BC_PERIODIC, BC_ODD):
        for kernel in (1, 2):
            CASES.append((scheme, 1, bc, kernel, 4))
            CASES.append((scheme, 1, bc, kernel, 8))


@pytest.mark.parametrize("scheme,dtype,bc,kernel,flags", CASES,
                         ids=lambda v: str(v))
@pytest.mark.parametrize("shape", [(13, 31), (130, 70)], ids=lambda s: f"{s[0]}x{s[1]}")
def test_section6_paths_keep_the_guard_band(w, scheme, dtype, bc, kernel, flags, shape):
    _exercise(w, scheme, dtype, bc, kernel, flags, shape)


@pytest.mark.parametrize("m", [28, 45])
@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("bc", [BC_ZERO, BC_PERIODIC, BC_ODD])
@pytest.mark.parametrize("kernel", [1, 2])
def test_derived_paths_keep_the_guard_band(w, m, dtype, bc, kernel):
    _exercise(w, w.derive_scheme(m), dtype, bc, kernel, 0, (150, 41))


@pytest.mark.parametrize("scheme", [5, 9, 13])
@pytest.mark.parametrize("kernel,T,rows", [(3, 4, 16), (3, 2, 32), (4, 4, 8), (4, 3, 37), (4, 4, 0)],
                         ids=["temporal-4-16", "temporal-2-32", "stream-4-8", "stream-3-37", "stream-4-auto"])
@pytest.mark.parametrize("shape", [(13, 31), (130, 70), (300, 97)], ids=lambda s: f"{s[0]}x{s[1]}")
def test_multilevel_kernels_keep_the_guard_band(w, scheme, kernel, T, rows, shape):
    """Zero boundary: the temporal kernels read ghost cells up to R T rows and
    16 columns out (canaries included, for nodes they force to zero) and must
    write inside the grid only; results equal a handle without canaries."""
    nx, ny = shape
    u0, v0, h = smooth_ic(nx, ny, BC_ZERO, seed=nx + T)
    lam = 0.5
    out = []
    for extra in (w.CANARY, 0):
        with w.Wave2D(nx, ny, h, lam * h, scheme=scheme, bc=BC_ZERO, dtype=w.F32, flags=extra) as sim:
            sim.set_tuning(kernel=kernel, temporal_t=T, tile_h=rows, use_graph=0)
            sim.first_step(u0, v0)
            sim.step_n(21)                                # T-level launches and single steps
            raw, k = sim.get_raw()
            sim.set_raw(raw, k)
            sim.set_tuning(kernel=kernel, temporal_t=T, tile_h=rows, use_graph=1)
            sim.step_n(40)                                # graph replays
            if extra:
                assert sim.canary_check() == 0
            out.append(sim.get_state())
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_canary_refusals(w):
    n = 64
    with w.Wave2D(n, n, 1.0 / n, 0.5 / n, scheme=13, dtype=w.F32, flags=w.CANARY) as sim:
        sim.set_tuning(kernel=w.KERNEL_STREAM)           # zero boundary: allowed
        with pytest.raises(w.Wave2DError) as e:
            w.Batch([sim])
        assert e.value.code == w.ERR_ARG
    with w.Wave2D(n, n, 1.0 / n, 0.5 / n, scheme=13, bc=BC_PERIODIC, dtype=w.F32, flags=w.CANARY) as sim:
        for kernel in (w.KERNEL_TEMPORAL, w.KERNEL_STREAM):
            with pytest.raises(w.Wave2DError) as e:
                sim.set_tuning(kernel=kernel)
            assert e.value.code == w.ERR_ARG
    with w.Wave2D(n, n, 1.0 / n, 0.5 / n, scheme=13, dtype=w.F32) as sim:
        with pytest.raises(w.Wave2DError) as e:
            sim.canary_check()
        assert e.value.code == w.ERR_STATE
