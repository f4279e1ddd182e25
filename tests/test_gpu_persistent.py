"""The persistent kernel (every level of a step_n call in one cooperative
launch, a grid barrier between levels): the same per-node arithmetic as the
one-node kernel, so its runs must equal single steps bit for bit for every
storage type, scheme and boundary, on ragged grids and grids larger than one
pass of the launch, across calls of any length and mode switches; plus parity
with the FP64 oracle and the bounded barrier wait (the self-test)."""
import numpy as np
import pytest

from gpu_util import TOL, rel_errors, smooth_ic
from initial_data import BC_PERIODIC, BC_ZERO, LAMBDA_MAX

pytestmark = pytest.mark.gpu

BC_ODD = 2


@pytest.fixture(scope="module")
def w():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1904_04048_gb300 import build
    build.build()
    from paper_1904_04048_gb300 import wave2d
    return wave2d


def run(w, scheme, dtype, bc, u0, v0, h, lam, chunks, tune):
    ny, nx = u0.shape
    with w.Wave2D(nx, ny, h, lam * h, scheme=scheme, bc=bc, dtype=dtype) as sim:
        sim.set_tuning(**tune)
        sim.first_step(u0, v0)
        for n in chunks:
            sim.step_n(n)
        up, uc, k = sim.get_state()
        raw, _ = sim.get_raw()
    return up, uc, k, raw


@pytest.mark.parametrize("dtype", [0, 1, 2], ids=["f64", "f32", "f32x2"])
@pytest.mark.parametrize("scheme", [5, 9, 13])
@pytest.mark.parametrize("bc", [BC_ZERO, BC_PERIODIC, BC_ODD], ids=["zero", "periodic", "odd"])
@pytest.mark.parametrize("shape", [(13, 31), (256, 256), (700, 333), (1, 40)], ids=lambda s: f"{s[0]}x{s[1]}")
def test_persistent_equals_single_steps_bitwise(w, dtype, scheme, bc, shape):
    nx, ny = shape
    u0, v0, h = smooth_ic(nx, ny, BC_ZERO if bc == BC_ODD else bc, seed=nx + 3 * ny + scheme)
    lam = 0.9 * LAMBDA_MAX[scheme]
    ref = run(w, scheme, dtype, bc, u0, v0, h, lam, [37], dict(kernel=w.KERNEL_SIMPLE, use_graph=0))
    got = run(w, scheme, dtype, bc, u0, v0, h, lam, [1, 0, 20, 16], dict(kernel=w.KERNEL_PERSISTENT))
    assert got[2] == ref[2] == 38
    assert np.array_equal(got[1], ref[1]) and np.array_equal(got[0], ref[0])
    assert np.array_equal(got[3], ref[3])  # every plane cell, ghost images included


def test_persistent_mode_switches_and_oracle(w, orc):
    n = 256
    u0, v0, h = smooth_ic(n, n, BC_ZERO, seed=2)
    lam = 0.5
    ref = run(w, 5, 0, BC_ZERO, u0, v0, h, lam, [199], dict(kernel=w.KERNEL_SIMPLE, use_graph=0))
    with w.Wave2D(n, n, h, lam * h, scheme=5, bc=BC_ZERO, dtype=0) as sim:
        sim.first_step(u0, v0)
        sim.set_tuning(kernel=w.KERNEL_PERSISTENT)
        sim.step_n(101)
        sim.set_tuning(kernel=w.KERNEL_TMA)
        sim.step_n(17)
        sim.set_tuning(kernel=w.KERNEL_PERSISTENT)
        sim.step_n(81)
        up, uc, k = sim.get_state()
    assert k == 200 and np.array_equal(uc, ref[1]) and np.array_equal(up, ref[0])
    rp, rc, _ = orc.run(5, u0, v0, lam, lam * h, 200, bc=BC_ZERO)
    for got, want in ((uc, rc), (up, rp)):
        l2, linf = rel_errors(got, want)
        assert l2 < TOL[0] and linf < TOL[0], (l2, linf)


def test_persistent_refuses_derived_and_difference_handles(w):
    s = w.derive_scheme(24)
    with w.Wave2D(64, 64, 1 / 64, 0.3 / 64, scheme=s, bc=BC_PERIODIC) as sim:
        with pytest.raises(w.Wave2DError) as e:
            sim.set_tuning(kernel=w.KERNEL_PERSISTENT)
        assert e.value.code == w.ERR_ARG
    with w.Wave2D(64, 64, 1 / 64, 0.3 / 64, scheme=13, bc=BC_PERIODIC, flags=w.DIFF_FORM) as sim:
        with pytest.raises(w.Wave2DError) as e:
            sim.set_tuning(kernel=w.KERNEL_PERSISTENT)
        assert e.value.code == w.ERR_ARG
