"""Batched stepping of many uneven simulations in one launch per quantum.

Each instance of a batch must end bit for bit where the same steps end on its
own handle (the per-node arithmetic is shared); checked for mixed sizes
(ragged, sub-tile and multi-tile), schemes, Courant numbers and step counts
(zero, and not multiples of the quantum), both boundaries, host and device
initial data, repeated runs (plan reuse), the batch autotuner's state
restoration, the batched norms, and against the FP64 oracle.
"""
import math

import numpy as np
import pytest

from gpu_util import TOL, rel_errors, smooth_ic
from initial_data import BC_PERIODIC, BC_ZERO, LAMBDA_MAX, batch_instances, instance_ic

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


def mixed_instances(bc, seed=0, count=14):
    rng = np.random.default_rng(seed)
    sizes = [(13, 31), (64, 64), (300, 97), (97, 300), (520, 75), (230, 230), (8, 8), (129, 65)]
    out = []
    for i in range(count):
        nx, ny = sizes[i % len(sizes)]
        scheme = [5, 9, 13][i % 3]
        lam = float(rng.uniform(0.3, 0.9 * LAMBDA_MAX[scheme]))
        steps = int(rng.integers(0, 60))
        u0, v0, h = smooth_ic(nx, ny, bc, seed=seed * 100 + i)
        out.append(dict(nx=nx, ny=ny, scheme=scheme, lam=lam, steps=steps, u0=u0, v0=v0, h=h))
    out[0]["steps"] = 0
    out[1]["steps"] = 4
    out[2]["steps"] = 61
    return out


def alone(w, inst, bc, steps_total):
    with w.Wave2D(inst["nx"], inst["ny"], inst["h"], inst["lam"] * inst["h"], scheme=inst["scheme"], bc=bc,
                  dtype=w.F32) as sim:
        sim.set_tuning(kernel=w.KERNEL_SIMPLE, use_graph=0)
        sim.first_step(inst["u0"], inst["v0"])
        sim.step_n(steps_total)
        return sim.get_state()


def make_handles(w, insts, bc):
    return [w.Wave2D(d["nx"], d["ny"], d["h"], d["lam"] * d["h"], scheme=d["scheme"], bc=bc, dtype=w.F32)
            for d in insts]


@pytest.mark.parametrize("bc", [BC_ZERO, BC_PERIODIC], ids=["zero", "periodic"])
@pytest.mark.parametrize("Tq,oh,kernel", [(4, 32, "regions"), (2, 64, "regions"), (3, 32, "regions"),
                                          (1, 32, "regions"), (4, 64, "stream"), (3, 16, "stream"),
                                          (2, 37, "stream"), (1, 8, "stream")])
def test_batch_equals_alone_bitwise(w, bc, Tq, oh, kernel):
    """Shared-memory regions (any boundary) and register streaming (zero
    boundary) end every instance where its own handle ends."""
    if kernel == "stream" and bc != BC_ZERO:
        pytest.skip("batched register streaming covers the zero boundary")
    kern = w.KERNEL_STREAM if kernel == "stream" else w.KERNEL_TEMPORAL
    insts = mixed_instances(bc, seed=Tq + oh)
    sims = make_handles(w, insts, bc)
    with w.Batch(sims, temporal_t=Tq, tile_h=oh, kernel=kern) as b:
        b.first_step([d["u0"] for d in insts], [d["v0"] for d in insts])
        b.run([d["steps"] for d in insts])
        for d, s in zip(insts, sims):
            up, uc, k = s.get_state()
            rp, rc, rk = alone(w, d, bc, d["steps"])
            assert k == rk == d["steps"] + 1
            assert np.array_equal(uc, rc) and np.array_equal(up, rp), (d["nx"], d["ny"], d["scheme"], d["steps"])
    for s in sims:
        s.close()


@pytest.mark.parametrize("bc", [BC_ZERO, BC_PERIODIC], ids=["zero", "periodic"])
def test_repeated_runs_and_device_inputs(w, bc):
    import torch
    insts = mixed_instances(bc, seed=9, count=9)
    sims = make_handles(w, insts, bc)
    with w.Batch(sims) as b:
        b.first_step([torch.from_numpy(d["u0"]).cuda() for d in insts],
                     [torch.from_numpy(d["v0"]).cuda() for d in insts])
        steps = [d["steps"] for d in insts]
        b.run(steps)
        b.run(steps)          # same counts: the captured run is replayed
        b.run([3] * len(insts))
        for d, s in zip(insts, sims):
            _, uc, k = s.get_state()
            _, rc, rk = alone(w, d, bc, 2 * d["steps"] + 3)
            assert k == rk and np.array_equal(uc, rc)
        # single-handle steps in between batch runs
        sims[3].step_n(5)
        b.run([2] * len(insts))
        _, uc, k = sims[3].get_state()
        _, rc, rk = alone(w, insts[3], bc, 2 * insts[3]["steps"] + 3 + 5 + 2)
        assert k == rk and np.array_equal(uc, rc)
    for s in sims:
        s.close()


def test_batch_norms_and_oracle_parity(w, orc):
    insts = mixed_instances(BC_ZERO, seed=4, count=6)
    sims = make_handles(w, insts, BC_ZERO)
    with w.Batch(sims) as b:
        b.first_step([d["u0"] for d in insts], [d["v0"] for d in insts])
        b.run([d["steps"] for d in insts])
        norms = b.norms()
    for d, s, (l2, mx) in zip(insts, sims, norms):
        ref_l2, ref_mx, _ = s.error_vs_exact()
        assert abs(l2 - ref_l2) <= 1e-12 * ref_l2 and mx == ref_mx
        _, uc, k = s.get_state()
        _, rc, _ = orc.run(d["scheme"], d["u0"], d["v0"], d["lam"], d["lam"] * d["h"], k, bc=BC_ZERO)
        l2e, linf = rel_errors(uc, rc)
        assert l2e < TOL[1] and linf < TOL[1]
    for s in sims:
        s.close()


def test_batch_autotune_restores_state(w):
    insts = mixed_instances(BC_PERIODIC, seed=11, count=8)
    sims = make_handles(w, insts, BC_PERIODIC)
    steps = [d["steps"] + 10 for d in insts]
    with w.Batch(sims) as b:
        b.first_step([d["u0"] for d in insts], [d["v0"] for d in insts])
        before = [s.get_state() for s in sims]
        best = b.autotune(steps, probe_steps=8)
        assert best.temporal_t in (2, 4) and best.tile_h in (32, 64)
        after = [s.get_state() for s in sims]
        for x, y in zip(before, after):
            assert x[2] == y[2] and np.array_equal(x[1], y[1]) and np.array_equal(x[0], y[0])
        b.run(steps)
        for d, s, n in zip(insts, sims, steps):
            _, uc, _ = s.get_state()
            _, rc, _ = alone(w, d, BC_PERIODIC, n)
            assert np.array_equal(uc, rc)
    for s in sims:
        s.close()


def test_batch_of_the_benchmark_distribution(w):
    """A sample of the mixed workload (log-uniform sizes, mixed schemes and
    step counts, centred pulses, zero boundary) against single handles."""
    insts = batch_instances(count=24, seed=4, steps_max=300)
    data = [instance_ic(i) for i in insts]
    sims = [w.Wave2D(i.n, i.n, h, i.lam * h, scheme=i.scheme, bc=BC_ZERO, dtype=w.F32)
            for i, (_, _, h) in zip(insts, data)]
    with w.Batch(sims) as b:
        b.first_step([d[0] for d in data], [d[1] for d in data])
        b.run([i.steps for i in insts])
        for i, (u0, v0, h), s in zip(insts, data, sims):
            _, uc, _ = s.get_state()
            ref = alone(w, dict(nx=i.n, ny=i.n, h=h, lam=i.lam, scheme=i.scheme, u0=u0, v0=v0), BC_ZERO, i.steps)
            assert np.array_equal(uc, ref[1])
    for s in sims:
        s.close()


def test_batch_argument_errors(w):
    a = w.Wave2D(16, 16, 0.1, 0.05, scheme=5, dtype=w.F64)
    b = w.Wave2D(16, 16, 0.1, 0.05, scheme=5, dtype=w.F32)
    c = w.Wave2D(16, 16, 0.1, 0.05, scheme=5, dtype=w.F32, bc=BC_PERIODIC)
    for bad in ([a], [b, c], [b, b]):
        with pytest.raises(w.Wave2DError) as e:
            w.Batch(bad)
        assert e.value.code == w.ERR_ARG
    with w.Batch([b]) as bb:
        with pytest.raises(w.Wave2DError) as e:
            bb.run([3])
        assert e.value.code == w.ERR_STATE
    for s in (a, b, c):
        s.close()


def test_stream_batch_reuse_direct_and_periodic_refusal(w):
    """Register-streaming batches: a repeated run replays its graph, direct
    launches (no graph) give the same bits, and a periodic batch is refused."""
    import ctypes
    insts = mixed_instances(BC_ZERO, seed=21, count=10)
    sims = make_handles(w, insts, BC_ZERO)
    steps = [d["steps"] for d in insts]
    with w.Batch(sims, kernel=w.KERNEL_STREAM, temporal_t=4, tile_h=32) as b:
        b.first_step([d["u0"] for d in insts], [d["v0"] for d in insts])
        b.run(steps)
        b.run(steps)
    # direct launches: wave2d_batch_create with use_graph = 0
    arr = (ctypes.c_void_p * len(sims))(*[s.handle.value for s in sims])
    opt = w.wave2d_tune(w.KERNEL_STREAM, 32, 4, 0, 0)
    bp = ctypes.c_void_p()
    w.check(w.lib().wave2d_batch_create(arr, len(sims), ctypes.byref(opt), ctypes.byref(bp)))
    try:
        st = (ctypes.c_int64 * len(sims))(*[3] * len(sims))
        w.check(w.lib().wave2d_batch_run(bp, st))
    finally:
        w.lib().wave2d_batch_destroy(bp)
    for d, s in zip(insts, sims):
        _, uc, k = s.get_state()
        _, rc, rk = alone(w, d, BC_ZERO, 2 * d["steps"] + 3)
        assert k == rk and np.array_equal(uc, rc)
    for s in sims:
        s.close()
    psims = make_handles(w, mixed_instances(BC_PERIODIC, seed=2, count=3), BC_PERIODIC)
    with pytest.raises(w.Wave2DError) as e:
        w.Batch(psims, kernel=w.KERNEL_STREAM)
    assert e.value.code == w.ERR_ARG
    for s in psims:
        s.close()


def test_zero_boundary_autotune_covers_streaming_and_restores(w):
    """On the zero boundary the batch autotuner also times register
    streaming; whatever it keeps, the state it timed on is restored and the
    run ends where single handles end."""
    insts = batch_instances(count=16, seed=4, steps_max=200)
    data = [instance_ic(i) for i in insts]
    sims = [w.Wave2D(i.n, i.n, h, i.lam * h, scheme=i.scheme, bc=BC_ZERO, dtype=w.F32)
            for i, (_, _, h) in zip(insts, data)]
    steps = [i.steps for i in insts]
    with w.Batch(sims) as b:
        b.first_step([d[0] for d in data], [d[1] for d in data])
        before = [s.get_state() for s in sims]
        best = b.autotune(steps, probe_steps=16)
        assert best.kernel in (w.KERNEL_TEMPORAL, w.KERNEL_STREAM) and 1 <= best.temporal_t <= 4
        after = [s.get_state() for s in sims]
        for x, y in zip(before, after):
            assert x[2] == y[2] and np.array_equal(x[1], y[1]) and np.array_equal(x[0], y[0])
        b.run(steps)
        for i, (u0, v0, h), s in zip(insts, data, sims):
            _, uc, _ = s.get_state()
            ref = alone(w, dict(nx=i.n, ny=i.n, h=h, lam=i.lam, scheme=i.scheme, u0=u0, v0=v0), BC_ZERO, i.steps)
            assert np.array_equal(uc, ref[1])
    for s in sims:
        s.close()
