"""The references of the plane-wave precision sweep (bench.py, precision leg)
against the oracle: at the sweep's full sizes and 10^4 steps, the runs the
sweep compares the other storage modes with — FP64 up to 2048^2, FP32x2
(double-float) at 4096^2 and 8192^2 — match the closed-form discrete
solution of Eq. A1 / A2 for a periodic plane wave (oracle/plane_wave.py,
itself pinned to the stepped FP64 oracle) on sampled nodes, to 1e-10.  The
longest and the shortest wave of the sweep are checked for the 9- and
13-point schemes."""
import math

import numpy as np
import pytest

from initial_data import BC_PERIODIC, LAMBDA_MAX, plane_wave_ic

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


@pytest.mark.parametrize("n,dtype", [(2048, 0), (4096, 2), (8192, 2)], ids=["2048-f64", "4096-f32x2", "8192-f32x2"])
@pytest.mark.parametrize("scheme", [9, 13])
@pytest.mark.parametrize("long_wave", [True, False], ids=["mode(1,0)", "mode(N/32,N/64)"])
def test_sweep_reference_matches_closed_form(w, n, dtype, scheme, long_wave):
    import torch
    from oracle import plane_wave
    import bench
    ref = [c for c in bench.precision_cases("bounded") if c[0] == n and c[1] == scheme]
    assert ref and ref[0][4] == {0: "f64", 2: "f32x2"}[dtype]     # the sweep's own reference
    m1, m2 = (1, 0) if long_wave else (n // 32, n // 64)
    steps = 10000
    h = 1.0 / n
    lam = 0.9 * LAMBDA_MAX[scheme]
    tau = lam * h
    k1, k2 = 2 * math.pi * m1, 2 * math.pi * m2
    u0, v0 = plane_wave_ic(n, n, h, k1, k2, BC_PERIODIC)
    du0, dv0 = torch.from_numpy(u0).cuda(), torch.from_numpy(v0).cuda()
    del u0, v0
    rng = np.random.default_rng(n + scheme)
    ii = rng.integers(0, n, 4096)
    jj = rng.integers(0, n, 4096)
    with w.Wave2D(n, n, h, tau, scheme=scheme, bc=BC_PERIODIC, dtype=dtype) as sim:
        sim.first_step(du0, dv0)
        sim.step_n(steps)
        shape, npdt = sim.row_block_shape(1)
        got = np.empty(len(ii))
        rows = {}
        for j in np.unique(jj):
            prev, cur = np.empty(shape, npdt), np.empty(shape, npdt)
            sim.get_rows(int(j), 1, prev, cur)
            rows[j] = cur.astype(np.float64).sum(axis=0) if dtype == 2 else cur[0]
        for q, (i, j) in enumerate(zip(ii, jj)):
            got[q] = rows[j].reshape(-1)[i]
        k = sim.info().k
    want = plane_wave.sample(scheme, lam, tau, k1, k2, h, k, ii, jj)
    err = np.max(np.abs(got - want)) / np.max(np.abs(want))
    assert err < 1e-10, err
