"""GPU parity of the derived schemes (segments M*_{<=m} beyond Section 6,
up to 41 stencil nodes, radius 4) through the C ABI.

* Every derived segment x storage type x boundary x kernel against the
  oracle's node-weight stepping (weights from its exact-rational
  derivation), on grids that span several tiles with ragged edges.
* The class-chain kernels with the 13-point coefficients reproduce the
  Section 6 kernels bit for bit; the TMA and one-node kernels agree bit for
  bit; results are D4-equivariant bit for bit.
* A full-size run (4096^2, 25 points) against the closed-form discrete
  plane wave; larger segments are more accurate against the PDE.
* Errors: instability, temporal kernel, batching and the conventional flag
  are refused for derived schemes.
"""
import math

import numpy as np
import pytest

from gpu_util import TOL, rel_errors, smooth_ic
from initial_data import BC_PERIODIC, BC_ZERO, plane_wave_ic
from oracle import derive, plane_wave

pytestmark = pytest.mark.gpu

DERIVED = (24, 28, 37, 41, 45)
SIZES = [(9, 11), (150, 77), (300, 70)]


@pytest.fixture(scope="module")
def w():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1904_04048_gb300 import build
    build.build()
    from paper_1904_04048_gb300 import wave2d
    return wave2d


def _lam(m):
    classes, a, _ = derive.class_scheme(m)
    return 0.9 * plane_wave.stability_limit(classes, lambda l: [derive.evaluate(p, l) for p in a])


def _run(w, scheme, u0, v0, h, lam, steps, bc, dtype, kernel):
    ny, nx = u0.shape
    with w.Wave2D(nx, ny, h, lam * h, scheme=scheme, bc=bc, dtype=dtype) as sim:
        sim.set_tuning(kernel=kernel, use_graph=0)
        sim.first_step(u0, v0)
        sim.step_n(steps - 1)
        up, uc, k = sim.get_state()
    assert k == steps
    return up, uc


@pytest.mark.parametrize("m", DERIVED)
@pytest.mark.parametrize("dtype,kernel", [(0, 1), (0, 2), (1, 1), (1, 2), (2, 1)],
                         ids=["f64-simple", "f64-tma", "f32-simple", "f32-tma", "f32x2-simple"])
@pytest.mark.parametrize("bc", [BC_ZERO, BC_PERIODIC], ids=["zero", "periodic"])
@pytest.mark.parametrize("shape", SIZES, ids=lambda s: f"{s[0]}x{s[1]}")
def test_parity_against_node_weight_oracle(orc, w, m, dtype, kernel, bc, shape):
    nx, ny = shape
    u0, v0, h = smooth_ic(nx, ny, bc, seed=m + nx)
    lam = _lam(m)
    steps = 30
    s = w.derive_scheme(m)
    up, uc = _run(w, s, u0, v0, h, lam, steps, bc, dtype, kernel)
    nodes, wa, wb = derive.node_weights(m, lam)
    rp, rc = orc.run_nodes(nodes, wa, wb, u0, v0, lam * h, steps, bc=bc)
    for got, ref in ((uc, rc), (up, rp)):
        l2, linf = rel_errors(got, ref)
        assert l2 < TOL[dtype] and linf < TOL[dtype], (l2, linf)


def _chain_copy_of_builtin(w, info, n_classes):
    """A scheme struct with constant coefficients equal to those a Section 6
    handle uses."""
    s = w.wave2d_scheme()
    s.segment, s.n_classes, s.radius, s.n_points = 0, n_classes, 0, 0
    for c in range(n_classes):
        s.a[c][0] = info.a[c]
        s.b[c][0] = info.b[c]
    return s


@pytest.mark.parametrize("scheme,nc", [(5, 1), (9, 2), (13, 3)])
@pytest.mark.parametrize("dtype,kernel", [(0, 1), (0, 2), (1, 1), (1, 2), (2, 1)])
def test_chain_kernels_reproduce_section6_kernels_bitwise(w, scheme, nc, dtype, kernel):
    n = 200
    u0, v0, h = smooth_ic(n, n - 37, BC_PERIODIC, seed=3)
    lam = 0.6
    out = []
    with w.Wave2D(n, n - 37, h, lam * h, scheme=scheme, bc=BC_PERIODIC, dtype=dtype) as ref:
        s = _chain_copy_of_builtin(w, ref.info(), nc)
        ref.set_tuning(kernel=kernel, use_graph=0)
        ref.first_step(u0, v0)
        ref.step_n(50)
        out.append(ref.get_raw()[0])
    with w.Wave2D(n, n - 37, h, lam * h, scheme=s, bc=BC_PERIODIC, dtype=dtype) as sim:
        sim.set_tuning(kernel=kernel, use_graph=0)
        sim.first_step(u0, v0)
        sim.step_n(50)
        out.append(sim.get_raw()[0])
    assert np.array_equal(out[0], out[1])


@pytest.mark.parametrize("m", [28, 45])
@pytest.mark.parametrize("dtype", [0, 1])
def test_tma_equals_simple_bitwise(w, m, dtype):
    n = 260
    u0, v0, h = smooth_ic(n, 150, BC_PERIODIC, seed=m)
    s = w.derive_scheme(m)
    lam = _lam(m)
    # the levels themselves (the TMA kernel also writes correct periodic
    # images of whole vectors a little beyond the R rings the readers use,
    # so the raw planes may differ in ghost cells nobody reads)
    states = []
    for kernel in (w.KERNEL_SIMPLE, w.KERNEL_TMA):
        with w.Wave2D(n, 150, h, lam * h, scheme=s, bc=BC_PERIODIC, dtype=dtype) as sim:
            sim.set_tuning(kernel=kernel, use_graph=0)
            sim.first_step(u0, v0)
            sim.step_n(60)
            states.append(sim.get_state())
    assert np.array_equal(states[0][0], states[1][0]) and np.array_equal(states[0][1], states[1][1])


@pytest.mark.parametrize("bc", [BC_ZERO, BC_PERIODIC])
@pytest.mark.parametrize("kernel", [1, 2])
def test_d4_symmetry_is_bitwise(w, bc, kernel):
    n = 133
    u0, v0, h = smooth_ic(n, n, bc, seed=11)
    s = w.derive_scheme(45)  # every class kind: four- and eight-node, radius 4
    lam = _lam(45)

    def run(a, b):
        with w.Wave2D(n, n, h, lam * h, scheme=s, bc=bc, dtype=1) as sim:
            sim.set_tuning(kernel=kernel, use_graph=0)
            sim.first_step(a, b)
            sim.step_n(40)
            return sim.get_state()[1]

    ref = run(u0, v0)
    for op in (lambda a: np.rot90(a).copy(), lambda a: a.T.copy(), lambda a: a[:, ::-1].copy()):
        assert np.array_equal(run(op(u0), op(v0)), op(ref))


def test_full_size_plane_wave_against_closed_form(w):
    """4096^2 periodic, 25-point scheme (m = 28), FP32 TMA kernel, 400 steps,
    sampled nodes against the closed-form discrete solution."""
    n, steps = 4096, 400
    h = 1.0 / n
    m = 28
    lam = _lam(m)
    tau = lam * h
    k1, k2 = 2 * math.pi * 3, 2 * math.pi * 4
    u0, v0 = plane_wave_ic(n, n, h, k1, k2, BC_PERIODIC)
    classes, a, b = derive.class_scheme(m)
    av = [derive.evaluate(p, lam) for p in a]
    bv = [derive.evaluate(p, lam) for p in b]
    with w.Wave2D(n, n, h, tau, scheme=w.derive_scheme(m), bc=BC_PERIODIC, dtype=1) as sim:
        sim.set_tuning(kernel=w.KERNEL_TMA)
        sim.first_step(u0, v0)
        sim.step_n(steps - 1)
        _, uc, _ = sim.get_state()
    rng = np.random.default_rng(7)
    ii, jj = rng.integers(0, n, 20000), rng.integers(0, n, 20000)
    an, bn = plane_wave.class_amplitudes(classes, av, bv, tau, k1, k2, h, steps)
    ph = k1 * ii * h + k2 * jj * h
    ref = an * np.cos(ph) + bn * np.sin(ph)
    got = uc[jj, ii]
    assert np.sqrt(np.mean((got - ref) ** 2)) / np.sqrt(np.mean(ref ** 2)) < 1e-5
    assert np.max(np.abs(got - ref)) < 1e-5


def test_larger_segments_are_more_accurate(w):
    """Against the PDE's plane wave, FP64, 256^2, lambda = 0.5: the error
    falls from the 13-point scheme through the derived 25- and 41-point
    schemes."""
    n = 256
    h = 1.0 / n
    k1, k2 = 2 * math.pi * 20, 2 * math.pi * 12
    u0, v0 = plane_wave_ic(n, n, h, k1, k2, BC_PERIODIC)
    lam, steps = 0.5, 400
    errs = []
    for scheme in (13, w.derive_scheme(28), w.derive_scheme(45)):
        with w.Wave2D(n, n, h, lam * h, scheme=scheme, bc=BC_PERIODIC, dtype=0) as sim:
            sim.first_step(u0, v0)
            sim.step_n(steps - 1)
            l2, _, _ = sim.error_vs_exact(w.exact(w.EXACT_PLANE, amp=1.0, k1=k1, k2=k2))
        errs.append(l2)
    # closed forms of the three schemes give 1.6e-2, 6.1e-4 and 2.5e-5
    assert errs[0] > 10 * errs[1] and errs[1] > 10 * errs[2], errs


def test_refusals(w):
    s = w.derive_scheme(24)
    lmax = w.scheme_lambda_max(s)
    n = 32
    with pytest.raises(w.Wave2DError) as e:
        w.Wave2D(n, n, 1.0 / n, 1.01 * lmax / n, scheme=s)
    assert e.value.code == w.ERR_UNSTABLE
    with pytest.raises(w.Wave2DError) as e:
        w.Wave2D(n, n, 1.0 / n, 0.5 / n, scheme=s, flags=w.CONVENTIONAL)
    assert e.value.code == w.ERR_ARG
    with w.Wave2D(n, n, 1.0 / n, 0.5 / n, scheme=s, dtype=1) as sim:
        with pytest.raises(w.Wave2DError) as e:
            sim.set_tuning(kernel=w.KERNEL_TEMPORAL)
        assert e.value.code == w.ERR_ARG
        inf = sim.info()
        assert inf.n_classes == 4 and inf.n_points == 21 and inf.radius == 2 and inf.scheme == 0
        with pytest.raises(w.Wave2DError) as e:
            w.Batch([sim])
        assert e.value.code == w.ERR_ARG
