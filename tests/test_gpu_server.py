"""Serving loop: continuous batching of independent simulations.

Requests of different sizes, schemes, Courant numbers and step counts are
submitted while others run; every result must equal the same request
computed alone (bit for bit for the levels, which share the per-node
arithmetic with a single handle), admission must respect the device-memory
budget and the slot limit, and invalid requests are refused at submission.
"""
import threading
import time

import numpy as np
import pytest

from gpu_util import TOL, rel_errors, smooth_ic
from initial_data import BC_ZERO, LAMBDA_MAX, gaussian_pulse

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


def requests(count=16, seed=0):
    rng = np.random.default_rng(seed)
    sizes = [(40, 40), (130, 70), (300, 97), (64, 200), (257, 257), (13, 31)]
    out = []
    for i in range(count):
        nx, ny = sizes[i % len(sizes)]
        scheme = [5, 9, 13][(i * 7) % 3]
        lam = float(rng.uniform(0.3, 0.9 * LAMBDA_MAX[scheme]))
        steps = int(rng.integers(0, 150))
        u0, v0, h = smooth_ic(nx, ny, BC_ZERO, seed=1000 + i)
        out.append(dict(tag=i, nx=nx, ny=ny, scheme=scheme, lam=lam, h=h, steps=steps, u0=u0, v0=v0))
    return out


def alone(w, r):
    with w.Wave2D(r["nx"], r["ny"], r["h"], r["lam"] * r["h"], scheme=r["scheme"], bc=BC_ZERO, dtype=w.F32) as s:
        s.set_tuning(kernel=w.KERNEL_SIMPLE, use_graph=0)
        s.first_step(r["u0"], r["v0"])
        s.step_n(r["steps"])
        _, uc, k = s.get_state()
        l2, linf, _ = s.error_vs_exact()
    return uc, k, l2, linf


def serve(w, reqs, stagger_s=0.0, **server_kw):
    outs = {r["tag"]: np.empty((r["ny"], r["nx"])) for r in reqs}
    comps = {}
    with w.Server(**server_kw) as srv:
        for r in reqs:
            srv.submit(r["nx"], r["ny"], r["h"], r["lam"] * r["h"], r["steps"], scheme=r["scheme"], u0=r["u0"],
                       v0=r["v0"], tag=r["tag"], out_field=outs[r["tag"]])
            if stagger_s:
                time.sleep(stagger_s)
        srv.drain(300)
        for c in srv.poll():
            comps[c.tag] = c
        st = srv.stats()
    return outs, comps, st


@pytest.mark.parametrize("quantum", [16, 64])
def test_results_in_the_mix_equal_alone(w, quantum):
    reqs = requests(16, seed=quantum)
    outs, comps, st = serve(w, reqs, stagger_s=0.002, quantum=quantum)
    assert st.completed == st.submitted == len(reqs)
    for r in reqs:
        c = comps[r["tag"]]
        assert c.status == 0
        uc, k, l2, linf = alone(w, r)
        assert c.k == k == r["steps"] + 1
        assert np.array_equal(outs[r["tag"]], uc), r["tag"]
        assert abs(c.l2 - l2) <= 1e-12 * l2 and c.linf == linf
        assert c.t_submit <= c.t_admit <= c.t_done


def test_single_request_server_equals_mixed_server(w):
    reqs = requests(10, seed=3)
    mixed, _, _ = serve(w, reqs)
    for r in reqs[:3]:
        solo, _, _ = serve(w, [r])
        assert np.array_equal(solo[r["tag"]], mixed[r["tag"]])


def test_budget_and_slots_limit_residency(w):
    reqs = requests(8, seed=5)
    biggest = max(w.lib().wave2d_required_bytes(r["nx"], r["ny"], w.F32) for r in reqs)
    outs, comps, st = serve(w, reqs, budget_bytes=biggest, quantum=32)
    assert st.completed == 8 and st.max_resident_seen == 1
    outs2, comps2, st2 = serve(w, reqs, max_resident=3, quantum=32)
    assert st2.completed == 8 and st2.max_resident_seen <= 3
    for r in reqs:
        assert np.array_equal(outs[r["tag"]], outs2[r["tag"]])


def test_concurrent_submitters_and_pulse_requests(w, orc):
    n, steps, scheme = 96, 120, 13
    h = 1.0 / (n + 1)
    lam = 0.6
    pulse = (1.0, 0.45, 0.55, 0.07)
    ref_u0 = gaussian_pulse(n, n, h, BC_ZERO, center=(0.45, 0.55), sigma=0.07)
    _, ref, _ = orc.run(scheme, ref_u0, np.zeros_like(ref_u0), lam, lam * h, steps + 1)
    outs = [np.empty((n, n)) for _ in range(12)]
    with w.Server(quantum=32) as srv:
        def submit(lo, hi):
            for t in range(lo, hi):
                srv.submit(n, n, h, lam * h, steps, scheme=scheme, pulse=pulse, tag=t, out_field=outs[t])
                time.sleep(0.001)
        th = [threading.Thread(target=submit, args=(6 * q, 6 * q + 6)) for q in range(2)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        srv.drain(300)
        comps = srv.poll()
    assert len(comps) == 12 and all(c.status == 0 for c in comps)
    for o in outs:
        assert np.array_equal(o, outs[0])
        l2, linf = rel_errors(o, ref)
        assert l2 < TOL[1] and linf < TOL[1]


def test_invalid_requests_are_refused(w):
    with w.Server(budget_bytes=64 << 20) as srv:
        with pytest.raises(w.Wave2DError) as e:
            srv.submit(64, 64, 0.1, 0.09, 10, scheme=5, pulse=(1, 0.5, 0.5, 0.1))  # lambda 0.9 > 1/sqrt2
        assert e.value.code == w.ERR_UNSTABLE
        with pytest.raises(w.Wave2DError) as e:
            srv.submit(8192, 8192, 1e-4, 5e-5, 10, scheme=5, pulse=(1, 0.5, 0.5, 0.1))
        assert e.value.code == w.ERR_OOM
        with pytest.raises(w.Wave2DError) as e:
            srv.submit(64, 64, 0.1, 0.05, 10, scheme=7, pulse=(1, 0.5, 0.5, 0.1))
        assert e.value.code == w.ERR_ARG
        srv.drain(10)


def test_staging_failure_fails_only_that_rounds_pulse_requests(w):
    """An allocator hook that refuses the initial-data staging of one pulse
    request (16 nx ny bytes): that request completes with WAVE2D_ERR_OOM and
    NaN norms, its levels are not counted, and a request served after it
    completes normally with the result it has alone."""
    import ctypes
    import torch
    nbad = 16 * 77 * 53                 # staging bytes of the 77 x 53 pulse request
    refused = []

    def _alloc(nbytes, stream, ctx):
        if int(nbytes) == nbad:
            refused.append(int(nbytes))
            return None
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), 0, int(stream or 0))
        except Exception:
            return None

    def _free(ptr, nbytes, stream, ctx):
        torch.cuda.caching_allocator_delete(int(ptr))

    refs = (w.ALLOC_FN(_alloc), w.FREE_FN(_free))
    w.check(w.lib().wave2d_set_allocator(refs[0], refs[1], None))
    try:
        h = 1.0 / 78
        with w.Server(budget_bytes=1 << 30, max_resident=8, quantum=16) as srv:
            srv.submit(77, 53, h, 0.5 * h, 40, scheme=13, pulse=(1.0, 0.5, 0.3, 0.1), tag=1)
            srv.drain(120)
            srv.submit(60, 60, h, 0.5 * h, 30, scheme=9, pulse=(1.0, 0.4, 0.4, 0.1), tag=2)
            srv.drain(120)
            comps = {int(c.tag): c for c in srv.poll(8)}
            st = srv.stats()
    finally:
        w.use_default_allocator()
    assert refused, "the hook never saw the staging allocation"
    bad, good = comps[1], comps[2]
    assert bad.status == w.ERR_OOM and np.isnan(bad.l2) and np.isnan(bad.linf)
    assert good.status == 0 and good.k == 31
    assert st.node_updates == 60 * 60 * 31           # the failed request's levels are not counted
    n = 60
    x = (np.arange(n) + 1) * h
    u0 = np.exp(-((x[None, :] - 0.4) ** 2 + (x[:, None] - 0.4) ** 2) / (2 * 0.1 ** 2))
    with w.Wave2D(n, n, h, 0.5 * h, scheme=9, bc=BC_ZERO, dtype=w.F32) as sim:
        sim.first_step(u0, np.zeros_like(u0))
        sim.step_n(30)
        l2, linf, _ = sim.error_vs_exact()
    assert abs(good.l2 - l2) <= 1e-6 * l2 and abs(good.linf - linf) <= 1e-6 * linf
