"""The class-chain modes on the register-streaming kernel, T levels per
launch, FP32:

* the difference form (WAVE2D_DIFF_FORM): d^{k+1} = d^k + Lambda_a(u^k),
  u^{k+1} = u^k + d^{k+1} (Eq. A2 on the pair u^k, d^k = u^k - u^{k-1});
* difference sums (WAVE2D_DIFF_SUMS): Eq. A2 with every class sum formed
  from differences to the centre;
* a derived scheme of three classes (13 points) with plain sums.

The per-node arithmetic is the one of the one-level kernels of each mode
(the same pairing and order), so the streamed levels equal the one-level
kernels' bit for bit: for the 5-, 9- and 13-point schemes, zero and periodic
boundaries, ragged shapes, every depth, strip heights, uneven runs (one-level
steps finish them), graph replays, raw state round trips and autotuning.
The one-level kernels themselves are pinned to the FP64 oracle in
test_gpu_diff_sums.py; here the streamed run is also checked against the
oracle and, for a long wave, against the closed-form discrete solution."""
import math

import numpy as np
import pytest

from gpu_util import TOL, rel_errors, smooth_ic
from initial_data import BC_PERIODIC, BC_ZERO, LAMBDA_MAX, plane_wave_ic
from oracle import plane_wave

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


def _run(w, scheme, u0, v0, h, lam, steps, bc, kernel, T=0, rows=0, graph=0, flags=None):
    ny, nx = u0.shape
    flags = w.DIFF_FORM if flags is None else flags
    with w.Wave2D(nx, ny, h, lam * h, scheme=scheme, bc=bc, dtype=w.F32, flags=flags) as sim:
        sim.set_tuning(kernel=kernel, temporal_t=T, tile_h=rows, use_graph=graph)
        if kernel == w.KERNEL_STREAM:
            assert sim.info().kernel == w.KERNEL_STREAM
        sim.first_step(u0, v0)
        sim.step_n(steps - 1)
        up, uc, k = sim.get_state()
        raw, _ = sim.get_raw()
        inf = sim.info()
    # d^k (difference form) or u^{k-1} as stored: the interior of the raw
    # state's first plane (its ghost ring holds periodic images that only the
    # kernels reading them refresh)
    g = inf.ghost
    d = np.frombuffer(raw.tobytes(), dtype=np.float32)[:inf.pitch * (ny + 2 * g)].reshape(ny + 2 * g, inf.pitch)
    return up, uc, k, d[g:g + ny, g:g + nx].copy()


def _same(a, b):
    return all(np.array_equal(x, y) for x, y in zip(a, b))


SHAPES = {BC_ZERO: [(13, 31), (300, 97), (257, 130)], BC_PERIODIC: [(300, 96), (132, 40), (16, 16)]}


@pytest.mark.parametrize("scheme", [5, 9, 13])
@pytest.mark.parametrize("bc", [BC_ZERO, BC_PERIODIC], ids=["zero", "periodic"])
@pytest.mark.parametrize("T", [2, 3, 4])
def test_stream_equals_one_level_bitwise(w, scheme, bc, T):
    lam = 0.9 * LAMBDA_MAX[scheme]
    for shape in SHAPES[bc]:
        nx, ny = shape
        u0, v0, h = smooth_ic(nx, ny, bc, seed=nx + 7 * scheme + T)
        ref = _run(w, scheme, u0, v0, h, lam, 43, bc, w.KERNEL_TMA)
        for rows in (16, 64):
            got = _run(w, scheme, u0, v0, h, lam, 43, bc, w.KERNEL_STREAM, T=T, rows=rows)
            assert got[2] == ref[2] == 43
            assert _same(got, ref), (shape, rows)


@pytest.mark.parametrize("scheme", [5, 9, 13])
@pytest.mark.parametrize("bc", [BC_ZERO, BC_PERIODIC], ids=["zero", "periodic"])
def test_stream_parity_with_oracle(orc, w, scheme, bc):
    nx, ny = (300, 96)
    u0, v0, h = smooth_ic(nx, ny, bc, seed=11 * scheme)
    lam = 0.9 * LAMBDA_MAX[scheme]
    steps = 40
    up, uc, k, _ = _run(w, scheme, u0, v0, h, lam, steps, bc, w.KERNEL_STREAM)
    rp, rc, _ = orc.run(scheme, u0, v0, lam, lam * h, steps, bc=bc)
    assert k == steps
    for got, ref in ((uc, rc), (up, rp)):
        l2, linf = rel_errors(got, ref)
        assert l2 < TOL[1] and linf < TOL[1], (l2, linf)


SUMS_SHAPES = {BC_ZERO: [(13, 31), (300, 97)], BC_PERIODIC: [(300, 96), (130, 41)]}


@pytest.mark.parametrize("scheme", [5, 9, 13])
@pytest.mark.parametrize("bc", [BC_ZERO, BC_PERIODIC], ids=["zero", "periodic"])
@pytest.mark.parametrize("T", [2, 3, 4, 6])
def test_difference_sums_stream_equals_one_level_bitwise(w, scheme, bc, T):
    """Periodic 130 x 41 takes the ghost-ring variant (rows not whole vectors)."""
    lam = 0.9 * LAMBDA_MAX[scheme]
    for nx, ny in SUMS_SHAPES[bc]:
        u0, v0, h = smooth_ic(nx, ny, bc, seed=nx + 5 * scheme + T)
        ref = _run(w, scheme, u0, v0, h, lam, 41, bc, w.KERNEL_TMA, flags=w.DIFF_SUMS)
        for rows in (16, 64):
            got = _run(w, scheme, u0, v0, h, lam, 41, bc, w.KERNEL_STREAM, T=T, rows=rows, flags=w.DIFF_SUMS)
            assert _same(got, ref), ((nx, ny), rows)


@pytest.mark.parametrize("flags", ["form", "sums", "plain"])
def test_derived_three_class_scheme_streams_bitwise(w, flags):
    s = w.derive_scheme(16)
    assert s.n_classes == 3
    fl = {"form": w.DIFF_FORM, "sums": w.DIFF_SUMS, "plain": 0}[flags]
    nx, ny = 260, 72
    lam = 0.9 * w.scheme_lambda_max(s)
    for bc in (BC_ZERO, BC_PERIODIC):
        u0, v0, h = smooth_ic(nx, ny, bc, seed=16)
        ref = _run(w, s, u0, v0, h, lam, 30, bc, w.KERNEL_TMA, flags=fl)
        for T in (3, 4):
            got = _run(w, s, u0, v0, h, lam, 30, bc, w.KERNEL_STREAM, T=T, rows=32, flags=fl)
            assert _same(got, ref), (bc, T)


def test_more_than_three_classes_do_not_stream(w):
    s = w.derive_scheme(28)
    assert s.n_classes > 3
    with w.Wave2D(256, 256, 1 / 256, 0.2 / 256, scheme=s, bc=BC_PERIODIC, dtype=w.F32) as sim:
        with pytest.raises(w.Wave2DError):
            sim.set_tuning(kernel=w.KERNEL_STREAM)


@pytest.mark.parametrize("scheme", [9, 13])
def test_graph_replays_equal_direct_launches(w, scheme):
    nx, ny = 256, 200
    for bc in (BC_ZERO, BC_PERIODIC):
        u0, v0, h = smooth_ic(nx, ny, bc, seed=scheme)
        lam = 0.8 * LAMBDA_MAX[scheme]
        a = _run(w, scheme, u0, v0, h, lam, 250, bc, w.KERNEL_STREAM, graph=0)
        b = _run(w, scheme, u0, v0, h, lam, 250, bc, w.KERNEL_STREAM, graph=1)
        c = _run(w, scheme, u0, v0, h, lam, 250, bc, w.KERNEL_TMA)
        assert _same(a, b) and _same(a, c)


def test_raw_round_trip_rows_and_autotune_keep_the_state(w):
    n = 320
    u0, v0, h = smooth_ic(n, n, BC_ZERO, seed=5)
    lam = 0.6
    with w.Wave2D(n, n, h, lam * h, scheme=13, bc=BC_ZERO, dtype=w.F32, flags=w.DIFF_FORM) as sim:
        sim.set_tuning(kernel=w.KERNEL_STREAM, temporal_t=3, use_graph=0)
        sim.first_step(u0, v0)
        sim.step_n(16)                      # odd number of launches: d^k sits in the second d plane
        raw, k = sim.get_raw()
        up0, uc0, _ = sim.get_state()
        best = sim.autotune(steps=12)       # state restored exactly
        assert sim.info().k == k and np.array_equal(sim.get_raw()[0], raw)
        assert best.kernel in (w.KERNEL_SIMPLE, w.KERNEL_TMA, w.KERNEL_STREAM)
        # rows out and back in: the state is unchanged
        import torch
        shape, _ = sim.row_block_shape(40)
        p = torch.empty(shape, dtype=torch.float32)
        c = torch.empty(shape, dtype=torch.float32)
        sim.get_rows(100, 40, p, c)        # difference form: d^k and u^k
        assert np.array_equal(c.numpy(), uc0[100:140].astype(np.float32))
        assert np.allclose(p.numpy(), uc0[100:140] - up0[100:140], rtol=0, atol=1e-7)
        sim.set_rows(100, 40, p, c)
        sim.set_tuning(kernel=w.KERNEL_STREAM, temporal_t=3, use_graph=0)
        sim.step_n(30)
        _, ref, _ = sim.get_state()
    with w.Wave2D(n, n, h, lam * h, scheme=13, bc=BC_ZERO, dtype=w.F32, flags=w.DIFF_FORM) as sim:
        sim.set_tuning(kernel=w.KERNEL_TMA, use_graph=0)
        sim.set_raw(raw, k)
        sim.step_n(30)
        _, got, kk = sim.get_state()
    assert kk == k + 30 and np.array_equal(got, ref)


def test_refusals(w):
    with w.Wave2D(130, 64, 1.0 / 130, 0.5 / 130, scheme=9, bc=BC_PERIODIC, dtype=w.F32, flags=w.DIFF_FORM) as sim:
        with pytest.raises(w.Wave2DError) as e:      # periodic rows not whole vectors
            sim.set_tuning(kernel=w.KERNEL_STREAM)
        assert e.value.code == w.ERR_ARG
    with w.Wave2D(128, 64, 1.0 / 128, 0.5 / 128, scheme=9, bc=BC_PERIODIC, dtype=w.F32, flags=w.DIFF_FORM) as sim:
        with pytest.raises(w.Wave2DError):
            sim.set_tuning(kernel=w.KERNEL_STREAM, temporal_t=6)
        with pytest.raises(w.Wave2DError):
            sim.set_tuning(kernel=w.KERNEL_TEMPORAL)
        sim.set_tuning(kernel=w.KERNEL_STREAM, temporal_t=4)
        assert sim.info().kernel == w.KERNEL_STREAM


@pytest.mark.parametrize("scheme", [9, 13])
def test_long_wave_accuracy_on_the_streaming_kernel(w, scheme):
    """Mode (1, 0), 1024^2 periodic, 3000 steps: the streamed difference form
    keeps the error against the closed-form discrete solution at least 20x
    below the plain two-step on the same kernel."""
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
        with w.Wave2D(n, n, h, tau, scheme=scheme, bc=BC_PERIODIC, dtype=w.F32, flags=flags) as sim:
            sim.set_tuning(kernel=w.KERNEL_STREAM, use_graph=0)
            sim.first_step(u0, v0)
            sim.step_n(steps - 1)
            _, uc, _ = sim.get_state()
        errs.append(float(np.sqrt(np.mean((uc - ref[None, :]) ** 2)) / np.sqrt(np.mean(ref ** 2))))
    assert errs[1] < errs[0] / 20, errs
