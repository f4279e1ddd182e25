"""Temporally blocked two-step (T levels per launch in shared memory).

Every node goes through the same per-node arithmetic as the one-step
kernels, so T steps of the temporal kernel must equal T single steps bit for
bit; these tests check that on ragged and tile-spanning grids, for both
boundaries, every scheme and every (T, tile height), across step counts that
are not multiples of T, mode switches in the middle of a run, CUDA-graph
replay and checkpoints; plus parity with the FP64 oracle and the autotuner's
exact restoration of the state it times on.
"""
import numpy as np
import pytest

from gpu_util import TOL, rel_errors, smooth_ic
from initial_data import BC_PERIODIC, BC_ZERO, LAMBDA_MAX

pytestmark = pytest.mark.gpu

SIZES = [(13, 31), (64, 64), (300, 97), (520, 75), (1000, 333)]


@pytest.fixture(scope="module")
def w():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1904_04048_gb300 import build
    build.build()
    from paper_1904_04048_gb300 import wave2d
    return wave2d


def run(w, scheme, u0, v0, h, lam, steps, bc, tune, chunks=None):
    ny, nx = u0.shape
    with w.Wave2D(nx, ny, h, lam * h, scheme=scheme, bc=bc, dtype=w.F32) as sim:
        sim.set_tuning(**tune)
        sim.first_step(u0, v0)
        for n in (chunks or [steps - 1]):
            sim.step_n(n)
        up, uc, k = sim.get_state()
    assert k == steps
    return up, uc


@pytest.mark.parametrize("scheme", [5, 9, 13])
@pytest.mark.parametrize("bc", [BC_ZERO, BC_PERIODIC], ids=["zero", "periodic"])
@pytest.mark.parametrize("T,oh", [(2, 32), (2, 64), (3, 24), (3, 32), (4, 16), (4, 24), (4, 32), (4, 64)])
@pytest.mark.parametrize("shape", SIZES, ids=lambda s: f"{s[0]}x{s[1]}")
def test_temporal_equals_single_steps_bitwise(w, scheme, bc, T, oh, shape):
    nx, ny = shape
    u0, v0, h = smooth_ic(nx, ny, bc, seed=nx + ny + T)
    lam = 0.9 * LAMBDA_MAX[scheme]
    steps = 38  # 37 two-steps: not a multiple of 2, 3 or 4
    ref = run(w, scheme, u0, v0, h, lam, steps, bc, dict(kernel=w.KERNEL_TMA, use_graph=0))
    got = run(w, scheme, u0, v0, h, lam, steps, bc,
              dict(kernel=w.KERNEL_TEMPORAL, temporal_t=T, tile_h=oh, use_graph=0))
    assert np.array_equal(got[1], ref[1]) and np.array_equal(got[0], ref[0])


@pytest.mark.parametrize("scheme", [5, 9, 13])
@pytest.mark.parametrize("bc", [BC_ZERO, BC_PERIODIC], ids=["zero", "periodic"])
@pytest.mark.parametrize("T,rows", [(2, 32), (3, 64), (4, 0), (4, 8), (4, 37), (4, 64), (4, 256), (6, 0), (6, 24),
                                    (6, 64)])
@pytest.mark.parametrize("shape", SIZES + [(5, 3), (121, 1), (1, 200)], ids=lambda s: f"{s[0]}x{s[1]}")
def test_stream_equals_single_steps_bitwise(w, scheme, bc, T, rows, shape):
    """The register-streaming kernel: strips of 128 columns (one warp) and
    8..256 rows, depths 2..6, grids from a single row or column to several
    strips each way with ragged edges."""
    nx, ny = shape
    u0, v0, h = smooth_ic(nx, ny, bc, seed=nx + ny + T + 1)
    lam = 0.9 * LAMBDA_MAX[scheme]
    steps = 38
    ref = run(w, scheme, u0, v0, h, lam, steps, bc, dict(kernel=w.KERNEL_TMA, use_graph=0))
    got = run(w, scheme, u0, v0, h, lam, steps, bc,
              dict(kernel=w.KERNEL_STREAM, temporal_t=T, tile_h=rows, use_graph=0))
    assert np.array_equal(got[1], ref[1]) and np.array_equal(got[0], ref[0])


@pytest.mark.parametrize("bc", [BC_ZERO, BC_PERIODIC], ids=["zero", "periodic"])
def test_stream_mode_switches_graphs_and_oracle(orc, w, bc):
    n = 260
    u0, v0, h = smooth_ic(n, n, bc, seed=15)
    lam = 0.6
    ref = run(w, 13, u0, v0, h, lam, 150, bc, dict(kernel=w.KERNEL_SIMPLE, use_graph=0))
    with w.Wave2D(n, n, h, lam * h, scheme=13, bc=bc, dtype=w.F32) as sim:
        sim.first_step(u0, v0)
        sim.set_tuning(kernel=w.KERNEL_STREAM, temporal_t=4, tile_h=64, use_graph=1)
        sim.step_n(70)          # a graph replay of 48 levels + 22 more
        assert sim.info().kernel == w.KERNEL_STREAM and sim.info().temporal_t == 4
        sim.set_tuning(kernel=w.KERNEL_TEMPORAL, temporal_t=4, use_graph=0)
        sim.step_n(21)
        sim.set_tuning(kernel=w.KERNEL_STREAM, temporal_t=3, tile_h=32, use_graph=0)
        sim.step_n(58)
        up, uc, k = sim.get_state()
    assert k == 150
    assert np.array_equal(uc, ref[1]) and np.array_equal(up, ref[0])
    rp, rc, _ = orc.run(13, u0, v0, lam, lam * h, 150, bc=bc)
    for got, want in ((uc, rc), (up, rp)):
        l2, linf = rel_errors(got, want)
        assert l2 < TOL[1] and linf < TOL[1], (l2, linf)


@pytest.mark.parametrize("scheme", [9, 13])
@pytest.mark.parametrize("bc", [BC_ZERO, BC_PERIODIC], ids=["zero", "periodic"])
def test_temporal_parity_with_oracle(orc, w, scheme, bc):
    nx, ny = 400, 210
    u0, v0, h = smooth_ic(nx, ny, bc, seed=77)
    lam = 0.9 * LAMBDA_MAX[scheme]
    up, uc = run(w, scheme, u0, v0, h, lam, 101, bc, dict(kernel=w.KERNEL_TEMPORAL, temporal_t=4))
    rp, rc, _ = orc.run(scheme, u0, v0, lam, lam * h, 101, bc=bc)
    for got, ref in ((uc, rc), (up, rp)):
        l2, linf = rel_errors(got, ref)
        assert l2 < TOL[1] and linf < TOL[1], (l2, linf)


@pytest.mark.parametrize("bc", [BC_ZERO, BC_PERIODIC], ids=["zero", "periodic"])
def test_mode_switches_and_graphs(w, bc):
    n = 260
    u0, v0, h = smooth_ic(n, n, bc, seed=5)
    lam = 0.6
    ref = run(w, 13, u0, v0, h, lam, 150, bc, dict(kernel=w.KERNEL_SIMPLE, use_graph=0))
    with w.Wave2D(n, n, h, lam * h, scheme=13, bc=bc, dtype=w.F32) as sim:
        sim.first_step(u0, v0)
        sim.set_tuning(kernel=w.KERNEL_TMA, use_graph=0)
        sim.step_n(21)
        sim.set_tuning(kernel=w.KERNEL_TEMPORAL, temporal_t=4, use_graph=1)
        sim.step_n(70)          # a graph replay of 48 levels + 22 more
        sim.set_tuning(kernel=w.KERNEL_SIMPLE, use_graph=0)
        sim.step_n(9)
        sim.set_tuning(kernel=w.KERNEL_TEMPORAL, temporal_t=2, tile_h=32, use_graph=0)
        sim.step_n(49)
        up, uc, k = sim.get_state()
    assert k == 150
    assert np.array_equal(uc, ref[1]) and np.array_equal(up, ref[0])


def test_temporal_checkpoint_resume(w):
    n = 300
    u0, v0, h = smooth_ic(n, n, BC_PERIODIC, seed=6)
    with w.Wave2D(n, n, h, 0.6 * h, scheme=9, bc=BC_PERIODIC, dtype=w.F32) as a:
        a.set_tuning(kernel=w.KERNEL_TEMPORAL, temporal_t=4)
        a.first_step(u0, v0)
        a.step_n(41)
        raw, k = a.get_raw()
        a.step_n(40)
        _, ref, _ = a.get_state()
    with w.Wave2D(n, n, h, 0.6 * h, scheme=9, bc=BC_PERIODIC, dtype=w.F32) as b:
        b.set_raw(raw, k)
        b.set_tuning(kernel=w.KERNEL_TEMPORAL, temporal_t=4)
        b.step_n(40)
        _, got, _ = b.get_state()
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("dtype", [0, 1])
def test_autotune_restores_state_and_keeps_results(w, dtype):
    n = 512
    u0, v0, h = smooth_ic(n, n, BC_PERIODIC, seed=8)
    with w.Wave2D(n, n, h, 0.6 * h, scheme=13, bc=BC_PERIODIC, dtype=dtype) as sim:
        sim.first_step(u0, v0)
        sim.step_n(10)
        before = sim.get_state()
        best = sim.autotune(steps=16)
        after = sim.get_state()
        assert after[2] == before[2] == 11
        assert np.array_equal(after[0], before[0]) and np.array_equal(after[1], before[1])
        assert best.kernel in (w.KERNEL_TMA, w.KERNEL_TEMPORAL, w.KERNEL_STREAM, w.KERNEL_SIMPLE)
        sim.step_n(30)
        _, got, _ = sim.get_state()
    with w.Wave2D(n, n, h, 0.6 * h, scheme=13, bc=BC_PERIODIC, dtype=dtype) as ref:
        ref.set_tuning(kernel=w.KERNEL_SIMPLE)
        ref.first_step(u0, v0)
        ref.step_n(40)
        _, want, _ = ref.get_state()
    assert np.array_equal(got, want)
