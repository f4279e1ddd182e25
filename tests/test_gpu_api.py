"""GPU behaviour of the C ABI: state and checkpoints, error codes, stability
guard, non-finite detection, CUDA-graph path, symmetry, allocator hook."""
import math

import numpy as np
import pytest

from gpu_util import TOL, rel_errors, smooth_ic
from initial_data import BC_PERIODIC, BC_ZERO, LAMBDA_MAX

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


def test_state_errors(w):
    with w.Wave2D(16, 16, 0.1, 0.05, scheme=5) as sim:
        with pytest.raises(w.Wave2DError) as e:
            sim.step_n(3)
        assert e.value.code == w.ERR_STATE
        with pytest.raises(w.Wave2DError) as e:
            sim.get_state()
        assert e.value.code == w.ERR_STATE
        sim.first_step(np.zeros((16, 16)), np.ones((16, 16)))
        with pytest.raises(w.Wave2DError) as e:
            sim.step_n(-1)
        assert e.value.code == w.ERR_ARG
        sim.step_n(0)
        assert sim.info().k == 1


@pytest.mark.parametrize("dtype", [0, 1, 2])
def test_checkpoint_resume_is_bitwise(w, dtype):
    n = 96
    u0, v0, h = smooth_ic(n, n, BC_PERIODIC, seed=1)
    lam = 0.6
    with w.Wave2D(n, n, h, lam * h, scheme=13, bc=BC_PERIODIC, dtype=dtype) as a:
        a.first_step(u0, v0)
        a.step_n(30)
        raw, k = a.get_raw()
        a.step_n(50)
        _, ref, _ = a.get_state()
    with w.Wave2D(n, n, h, lam * h, scheme=13, bc=BC_PERIODIC, dtype=dtype) as b:
        b.set_raw(raw, k)
        b.step_n(50)
        _, got, kk = b.get_state()
    assert kk == 81 and np.array_equal(got, ref)


@pytest.mark.parametrize("dtype", [0, 1])
def test_set_state_resumes(w, orc, dtype):
    n = 50
    u0, v0, h = smooth_ic(n, n, BC_ZERO, seed=2)
    lam = 0.5
    rp, rc, _ = orc.run(9, u0, v0, lam, lam * h, 10, bc=BC_ZERO)
    with w.Wave2D(n, n, h, lam * h, scheme=9, bc=BC_ZERO, dtype=dtype) as sim:
        sim.set_state(rp, rc, 10)
        sim.step_n(20)
        _, got, k = sim.get_state()
    _, ref = orc.continue_run(9, rp, rc, lam, 20, bc=BC_ZERO)
    assert k == 30
    l2, linf = rel_errors(got, ref)
    assert l2 < TOL[dtype] and linf < TOL[dtype]


def test_graph_path_is_bitwise_equal(w):
    n = 200
    u0, v0, h = smooth_ic(n, n, BC_PERIODIC, seed=4)
    out = []
    for use_graph in (0, 1):
        with w.Wave2D(n, n, h, 0.6 * h, scheme=13, bc=BC_PERIODIC, dtype=1) as sim:
            sim.set_tuning(kernel=w.KERNEL_TMA, use_graph=use_graph)
            sim.first_step(u0, v0)
            sim.step_n(101)  # 3 graph replays of 32 steps + 5 single launches
            out.append(sim.get_state())
    assert out[0][2] == out[1][2] == 102
    assert np.array_equal(out[0][1], out[1][1]) and np.array_equal(out[0][0], out[1][0])


@pytest.mark.parametrize("bc", [BC_ZERO, BC_PERIODIC])
@pytest.mark.parametrize("kernel", [1, 2])
def test_d4_symmetry_is_bitwise(w, bc, kernel):
    """Each stencil sum pairs opposite neighbours, so rotating or reflecting
    the data permutes operands of commutative additions only."""
    n = 131
    u0, v0, h = smooth_ic(n, n, bc, seed=9)
    def run(a, b):
        with w.Wave2D(n, n, h, 0.6 * h, scheme=13, bc=bc, dtype=1) as sim:
            sim.set_tuning(kernel=kernel)
            sim.first_step(a, b)
            sim.step_n(60)
            return sim.get_state()[1]
    ref = run(u0, v0)
    for op in (lambda a: np.rot90(a).copy(), lambda a: a.T.copy(), lambda a: a[::-1].copy()):
        assert np.array_equal(run(op(u0), op(v0)), op(ref))


def test_instability_and_nonfinite_detection(w):
    n = 64
    rng = np.random.default_rng(0)
    u0 = rng.standard_normal((n, n))
    v0 = rng.standard_normal((n, n))
    h = 1.0 / n
    lam = 1.5 * LAMBDA_MAX[13]
    with pytest.raises(w.Wave2DError) as e:
        w.Wave2D(n, n, h, lam * h, scheme=13)
    assert e.value.code == w.ERR_UNSTABLE
    with w.Wave2D(n, n, h, lam * h, scheme=13, bc=BC_PERIODIC, dtype=1, flags=w.ALLOW_UNSTABLE) as sim:
        sim.first_step(u0, v0)
        sim.step_n(20)
        l2, linf, _ = sim.error_vs_exact()
        assert np.isfinite(l2) and l2 > 1e3
        sim.step_n(2000)
        with pytest.raises(w.Wave2DError) as e:
            sim.error_vs_exact()
        assert e.value.code == w.ERR_NONFINITE


def test_stability_edge_is_accepted(w):
    for scheme in (5, 9, 13):
        lm = w.lambda_max(scheme)
        with w.Wave2D(8, 8, 1.0, lm, scheme=scheme):
            pass


def test_device_inputs_and_torch_allocator(w, orc):
    import torch
    n = 80
    u0, v0, h = smooth_ic(n, n, BC_ZERO, seed=6)
    w.use_torch_allocator()
    try:
        with w.Wave2D(n, n, h, 0.5 * h, scheme=5, dtype=0) as sim:
            sim.first_step(torch.from_numpy(u0).cuda(), torch.from_numpy(v0).cuda())
            sim.step_n(25)
            _, got, _ = sim.get_state()
    finally:
        w.use_default_allocator()
    _, ref, _ = orc.run(5, u0, v0, 0.5, 0.5 * h, 26)
    l2, linf = rel_errors(got, ref)
    assert l2 < 1e-12 and linf < 1e-12


def test_user_stream(w):
    import torch
    s = torch.cuda.Stream()
    n = 64
    u0, v0, h = smooth_ic(n, n, BC_PERIODIC, seed=8)
    with w.Wave2D(n, n, h, 0.5 * h, scheme=9, bc=BC_PERIODIC, stream=s.cuda_stream) as sim:
        sim.first_step(u0, v0)
        sim.step_n(10)
        sim.sync()
        assert sim.info().k == 11


def test_launch_counter_counts_kernels(w):
    n = 64
    u0, v0, h = smooth_ic(n, n, BC_PERIODIC, seed=8)
    with w.Wave2D(n, n, h, 0.5 * h, scheme=9, bc=BC_PERIODIC) as sim:
        sim.set_tuning(kernel=w.KERNEL_SIMPLE, use_graph=0)
        sim.first_step(u0, v0)
        c0 = w.launch_count()
        sim.step_n(17)
        assert w.launch_count() - c0 == 17


def test_bounded_wait_times_out_and_reports(w):
    """A wait that nothing completes gives up after its limit; the host reads
    WAVE2D_ERR_TIMEOUT at the next synchronising call, the status is cleared
    and the handle keeps working."""
    n = 64
    u0, v0, h = smooth_ic(n, n, BC_PERIODIC, seed=3)
    with w.Wave2D(n, n, h, 0.5 * h, scheme=13, bc=BC_PERIODIC, dtype=w.F32) as sim:
        sim.first_step(u0, v0)
        sim.selftest_timeout(1 << 20)  # about 0.5 ms of SM clocks
        with pytest.raises(w.Wave2DError) as e:
            sim.sync()
        assert e.value.code == w.ERR_TIMEOUT
        sim.sync()  # cleared
        sim.step_n(5)
        _, uc, k = sim.get_state()
        assert k == 6 and np.all(np.isfinite(uc))


def test_temporal_tuning_is_validated(w):
    n = 64
    with w.Wave2D(n, n, 1.0 / n, 0.5 / n, scheme=13, bc=BC_PERIODIC, dtype=w.F32) as sim:
        for bad in (dict(temporal_t=1), dict(temporal_t=8), dict(tile_h=40), dict(tile_h=-1)):
            with pytest.raises(w.Wave2DError) as e:
                sim.set_tuning(kernel=w.KERNEL_TEMPORAL, **bad)
            assert e.value.code == w.ERR_ARG
        for oh in (16, 24, 32, 64):
            sim.set_tuning(kernel=w.KERNEL_TEMPORAL, temporal_t=2, tile_h=oh)
            assert sim.info().temporal_t == 2


def test_stream_tuning_is_validated(w):
    n = 64
    with w.Wave2D(n, n, 1.0 / n, 0.5 / n, scheme=9, bc=BC_PERIODIC, dtype=w.F32) as sim:
        for bad in (dict(temporal_t=1), dict(temporal_t=5), dict(tile_h=7), dict(tile_h=4097), dict(tile_h=-1)):
            with pytest.raises(w.Wave2DError) as e:
                sim.set_tuning(kernel=w.KERNEL_STREAM, **bad)
            assert e.value.code == w.ERR_ARG
        with pytest.raises(w.Wave2DError) as e:
            sim.set_tuning(kernel=6)   # no such kernel
        assert e.value.code == w.ERR_ARG
        for rows in (0, 8, 37, 4096):
            sim.set_tuning(kernel=w.KERNEL_STREAM, temporal_t=3, tile_h=rows)
            assert sim.info().kernel == w.KERNEL_STREAM and sim.info().temporal_t == 3
    with w.Wave2D(n, n, 1.0 / n, 0.5 / n, scheme=9, bc=BC_PERIODIC, dtype=w.F64) as sim:
        sim.set_tuning(kernel=w.KERNEL_STREAM)   # FP64: falls back to a one-level kernel
        assert sim.info().kernel in (w.KERNEL_TMA, w.KERNEL_SIMPLE)


def test_alu_peaks_are_measured_rates(w):
    """wave2d_alu_peaks: FP32 lane-operation rates within [0.5, 1.2] of the
    device's 128 FP32 lanes per SM at its clock attribute, and FP64 well
    below FP32 (GB300's FP64 rate is a small fraction of its FP32 rate)."""
    p = w.alu_peaks()
    assert p.sms > 0 and p.clock_khz > 0
    spec = p.sms * 128 * p.clock_khz * 1e3
    for v in (p.fp32_fma, p.fp32_fma2, p.fp32_add):
        assert 0.5 * spec < v < 1.2 * spec, (v, spec)
    assert 0 < p.fp64_fma < 0.5 * p.fp32_fma


def test_diff_norms_match_the_host_difference(w):
    """wave2d_diff_norms: the FP64 norms of the difference of two handles'
    current levels, relative to the second, equal the host computation from
    the two states; mismatched sizes or levels are refused."""
    import math as _m
    n = 96
    h = 1.0 / n
    k1, k2 = 2 * _m.pi * 3, 2 * _m.pi * 1
    from initial_data import plane_wave_ic
    u0, v0 = plane_wave_ic(n, n, h, k1, k2, BC_PERIODIC)
    with w.Wave2D(n, n, h, 0.5 * h, scheme=13, bc=BC_PERIODIC, dtype=w.F32) as a, \
            w.Wave2D(n, n, h, 0.5 * h, scheme=13, bc=BC_PERIODIC, dtype=w.F64) as b, \
            w.Wave2D(n, n + 1, h, 0.5 * h, scheme=13, bc=BC_PERIODIC, dtype=w.F64) as c:
        for sim in (a, b):
            sim.first_step(u0, v0)
            sim.step_n(300)
        l2, linf = a.diff_norms(b)
        _, ua, _ = a.get_state()
        _, ub, _ = b.get_state()
        d = ua - ub
        assert abs(l2 - np.linalg.norm(d) / np.linalg.norm(ub)) <= 1e-12 * l2
        assert abs(linf - np.max(np.abs(d)) / np.max(np.abs(ub))) <= 1e-12 * linf
        assert 1e-9 < l2 < 1e-4                       # FP32 rounding, not zero
        assert b.diff_norms(b) == (0.0, 0.0)
        with pytest.raises(w.Wave2DError) as e:       # different grid
            c.first_step(np.zeros((n + 1, n)), np.zeros((n + 1, n)))
            a.diff_norms(c)
        assert e.value.code == w.ERR_ARG
        a.step_n(1)
        with pytest.raises(w.Wave2DError) as e:       # different level
            a.diff_norms(b)
        assert e.value.code == w.ERR_STATE
