"""Parity at the full benchmark size, in the launch configuration the
benchmark times (FP32 storage, 4096^2 periodic grid, lambda = 0.9 lambda_max,
9- and 13-point schemes; the automatic kernel, which is the register-streaming
kernel at this size, the streaming kernel with the strip heights bench.py
--fixed-tuning pins, and the shared-memory temporal kernel the autotuner may
choose instead).

* Multi-pulse displacement plus band-limited velocity (the benchmark's
  inputs): the whole field after 10 steps against the FP64 oracle run at the
  same size.
* Periodic plane wave for the benchmark's 2000 steps: the whole field against
  the closed-form discrete solution (exact at any size).
"""
import math

import numpy as np
import pytest

from gpu_util import rel_errors
from initial_data import BC_PERIODIC, LAMBDA_MAX, plane_wave_ic, pulses_and_noise

pytestmark = pytest.mark.gpu
N = 4096


@pytest.fixture(scope="module")
def w():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1904_04048_gb300 import build
    build.build()
    from paper_1904_04048_gb300 import wave2d
    return wave2d


@pytest.fixture(scope="module")
def bench_ic():
    return pulses_and_noise(N, seed=2019)


@pytest.mark.parametrize("scheme", [9, 13])
@pytest.mark.parametrize("kernel", ["auto", "temporal", "bench-fixed"])
def test_benchmark_inputs_against_oracle(w, orc, bench_ic, scheme, kernel):
    u0, v0 = bench_ic
    h = 1.0 / N
    lam = 0.9 * LAMBDA_MAX[scheme]
    steps = 10
    with w.Wave2D(N, N, h, lam * h, scheme=scheme, bc=BC_PERIODIC, dtype=1) as sim:
        if kernel == "auto":
            assert sim.info().kernel == w.KERNEL_STREAM  # automatic choice at this size
        elif kernel == "temporal":
            sim.set_tuning(kernel=w.KERNEL_TEMPORAL, temporal_t=4)
        else:  # the strips bench.py --fixed-tuning pins (the autotuner's usual choice)
            from bench import FIXED_TUNING
            name, rows, depth = FIXED_TUNING[scheme]
            assert name == "stream"
            sim.set_tuning(kernel=w.KERNEL_STREAM, temporal_t=depth, tile_h=rows)
            assert sim.info().kernel == w.KERNEL_STREAM
        sim.first_step(u0, v0)
        sim.step_n(steps - 1)
        up, uc, _ = sim.get_state()
    rp, rc, _ = orc.run(scheme, u0, v0, lam, lam * h, steps, bc=BC_PERIODIC)
    for got, ref in ((uc, rc), (up, rp)):
        l2, linf = rel_errors(got, ref)
        assert l2 < 1e-6 and linf < 1e-6, (l2, linf)


@pytest.mark.parametrize("scheme", [9, 13])
def test_plane_wave_2000_steps_against_closed_form(w, scheme):
    from oracle import plane_wave
    h = 1.0 / N
    lam = 0.9 * LAMBDA_MAX[scheme]
    tau = lam * h
    k1, k2 = 2 * math.pi * (N // 32), 2 * math.pi * (N // 64)
    u0, v0 = plane_wave_ic(N, N, h, k1, k2, BC_PERIODIC)
    steps = 2000
    with w.Wave2D(N, N, h, tau, scheme=scheme, bc=BC_PERIODIC, dtype=1) as sim:
        sim.first_step(u0, v0)
        sim.step_n(steps - 1)
        _, uc, _ = sim.get_state()
    ref = plane_wave.field(scheme, lam, tau, k1, k2, h, N, N, steps)
    l2, linf = rel_errors(uc, ref)
    # FP32 bound: 1e-5 per 1000 steps (storage and coefficient rounding both
    # accumulate linearly in the phase).
    assert l2 < 2e-5 and linf < 2e-5, (l2, linf)
